// scene.cu - scene upload, validation and packing into the device layout;
// error reporting of the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "nrc_internal.cuh"
#include "rtb_internal.cuh"

namespace rtb {

static thread_local std::string g_last_error;

rt_status set_error(rt_status st, const std::string& msg) {
  if (st != RT_OK) g_last_error = msg;
  return st;
}

rt_status cuda_error(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return RT_OK;
  cudaGetLastError();  // clear the sticky-free error state
  return set_error(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

rt_status ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.p && b.bytes >= bytes) return RT_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc");
  b.bytes = bytes;
  ++b.gen;
  return RT_OK;
}

void release(Buf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// One thread per primitive: ABI structs -> 48-byte records (primitive-id
// order).  Edges are formed once here, in FP32.  A material index out of
// range (possible only through rt_scene_update) becomes 0 and is reported.
__global__ void k_pack(const rt_sphere* __restrict__ sph, int ns, const rt_triangle* __restrict__ tri, int nt,
                       uint32_t n_mats, float4* __restrict__ out, unsigned* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns + nt) return;
  float4 r0, r1, r2;
  uint32_t mat;
  if (i < ns) {
    const rt_sphere& s = sph[i];
    float r = s.radius;
    mat = s.material;
    r0 = make_float4(s.center[0], s.center[1], s.center[2], __int_as_float(kKindSphere));
    r1 = make_float4(r, r * r, 0.f, __int_as_float(i));
    r2 = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    const rt_triangle& t = tri[i - ns];
    float v0x = t.v0[0], v0y = t.v0[1], v0z = t.v0[2];
    mat = t.material;
    r0 = make_float4(v0x, v0y, v0z, __int_as_float(kKindTriangle));
    r1 = make_float4(t.v1[0] - v0x, t.v1[1] - v0y, t.v1[2] - v0z, __int_as_float(i));
    r2 = make_float4(t.v2[0] - v0x, t.v2[1] - v0y, t.v2[2] - v0z, 0.f);
  }
  if (mat >= n_mats) {
    atomicOr(status, kErrBadMaterial);
    mat = 0;
  }
  r2.w = __int_as_float((int)mat);
  out[3 * (size_t)i + 0] = r0;
  out[3 * (size_t)i + 1] = r1;
  out[3 * (size_t)i + 2] = r2;
}

static rt_status pack(rt_scene* s, cudaStream_t st) {
  int n = (int)s->n_prims;
  if (n == 0) return RT_OK;
  k_pack<<<(n + 255) / 256, 256, 0, st>>>((const rt_sphere*)s->raw_sph.p, (int)s->n_spheres,
                                          (const rt_triangle*)s->raw_tri.p, (int)s->n_tris,
                                          (uint32_t)s->n_mats, (float4*)s->prims_id.p, s->status);
  return cuda_error(cudaGetLastError(), "k_pack");
}

static float bits_as_float(int v) {
  float f;
  memcpy(&f, &v, sizeof f);
  return f;
}

static bool finite3(const float* p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

DevScene dev_scene(const rt_scene* s, bool use_bvh) {
  DevScene d;
  d.prims = (const float4*)(use_bvh ? s->prims_leaf.p : s->prims_id.p);
  d.nodes = (const float4*)s->nodes4.p;
  d.mats = (const float4*)s->mats.p;
  d.lights = (const float4*)s->lights.p;
  d.n_prims = (int)s->n_prims;
  d.n_lights = (int)s->n_lights;
  d.alights = (const float4*)s->alights.p;
  d.n_alights = (int)s->n_alights;
  d.prims_id = (const float4*)s->prims_id.p;
  d.emitters = (const int*)s->emitters.p;
  d.n_emitters = (int)s->n_emitters;
  d.n_nodes = (int)s->n_nodes4;
  d.root = use_bvh ? s->root : -1;
  d.use_bvh = use_bvh ? 1 : 0;
  d.traversal_cap = 0;
  d.status = s->status;
  return d;
}

}  // namespace rtb

using namespace rtb;

extern "C" {

int rt_abi_version(void) { return RTB_ABI_VERSION; }

const char* rt_last_error(void) { return g_last_error.c_str(); }

void rt_render_options_default(rt_render_options* o) {
  if (!o) return;
  o->use_bvh = 1;
  o->flags = 0;
  o->background[0] = o->background[1] = o->background[2] = 0.1f;
  o->eps_scale = 1e-4f;
  o->queue_capacity = 0;
  o->traversal_cap = 0;
  o->ray_counts = nullptr;
}

rt_status rt_scene_create(const rt_sphere* spheres, size_t n_spheres, const rt_triangle* triangles,
                          size_t n_triangles, const rt_material* materials, size_t n_materials,
                          const rt_point_light* lights, size_t n_lights, rt_scene** out) {
  if (!out) return set_error(RT_ERR_INVALID_ARG, "rt_scene_create: out is NULL");
  *out = nullptr;
  if ((n_spheres && !spheres) || (n_triangles && !triangles) || (n_lights && !lights))
    return set_error(RT_ERR_INVALID_ARG, "rt_scene_create: NULL array with a non-zero count");
  if (!materials || n_materials == 0)
    return set_error(RT_ERR_INVALID_ARG, "rt_scene_create: at least one material is required");
  if (n_spheres + n_triangles >= (size_t)1 << 28)
    return set_error(RT_ERR_UNSUPPORTED, "rt_scene_create: more than 2^28 primitives");
  for (size_t i = 0; i < n_spheres; ++i) {
    const rt_sphere& s = spheres[i];
    if (!finite3(s.center) || !std::isfinite(s.radius))
      return set_error(RT_ERR_INVALID_ARG, "sphere " + std::to_string(i) + ": non-finite value");
    if (!(s.radius > 0.f)) return set_error(RT_ERR_INVALID_ARG, "sphere " + std::to_string(i) + ": radius <= 0");
    if (s.material >= n_materials)
      return set_error(RT_ERR_INVALID_ARG, "sphere " + std::to_string(i) + ": material index out of range");
  }
  for (size_t i = 0; i < n_triangles; ++i) {
    const rt_triangle& t = triangles[i];
    if (!finite3(t.v0) || !finite3(t.v1) || !finite3(t.v2))
      return set_error(RT_ERR_INVALID_ARG, "triangle " + std::to_string(i) + ": non-finite vertex");
    if (t.material >= n_materials)
      return set_error(RT_ERR_INVALID_ARG, "triangle " + std::to_string(i) + ": material index out of range");
  }
  for (size_t i = 0; i < n_materials; ++i) {
    const rt_material& m = materials[i];
    bool ok = finite3(m.albedo) && finite3(m.emission) && std::isfinite(m.ks) && std::isfinite(m.shininess) &&
              std::isfinite(m.reflectivity) && std::isfinite(m.ior) && m.kind <= RT_MAT_DIELECTRIC;
    if (ok && m.kind == RT_MAT_DIELECTRIC && !(m.ior > 0.f)) ok = false;
    if (!ok) return set_error(RT_ERR_INVALID_ARG, "material " + std::to_string(i) + ": invalid");
  }
  for (size_t i = 0; i < n_lights; ++i)
    if (!finite3(lights[i].position) || !finite3(lights[i].intensity))
      return set_error(RT_ERR_INVALID_ARG, "light " + std::to_string(i) + ": non-finite value");

  rt_scene* s = new rt_scene();
  {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (size_t i = 0; i < n_spheres; ++i)
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], spheres[i].center[k] - spheres[i].radius);
        hi[k] = std::max(hi[k], spheres[i].center[k] + spheres[i].radius);
      }
    for (size_t i = 0; i < n_triangles; ++i)
      for (int k = 0; k < 3; ++k) {
        const rt_triangle& t = triangles[i];
        lo[k] = std::min(lo[k], std::min(t.v0[k], std::min(t.v1[k], t.v2[k])));
        hi[k] = std::max(hi[k], std::max(t.v0[k], std::max(t.v1[k], t.v2[k])));
      }
    for (int k = 0; k < 3; ++k)
      if (lo[k] <= hi[k]) {
        s->bbox_lo[k] = lo[k];
        s->bbox_hi[k] = hi[k];
      }
  }
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  preload_frame_kernels(s->device);
  s->n_spheres = (int64_t)n_spheres;
  s->n_tris = (int64_t)n_triangles;
  s->n_prims = s->n_spheres + s->n_tris;
  s->n_mats = (int64_t)n_materials;
  s->n_lights = (int64_t)n_lights;
  rt_status st = RT_OK;
  std::vector<float4> mats(3 * n_materials), lts(2 * (n_lights ? n_lights : 1));
  for (size_t i = 0; i < n_materials; ++i) {
    const rt_material& m = materials[i];
    mats[3 * i + 0] = make_float4(m.albedo[0], m.albedo[1], m.albedo[2], m.ks);
    mats[3 * i + 1] = make_float4(m.shininess, m.reflectivity, m.ior, bits_as_float((int)m.kind));
    mats[3 * i + 2] = make_float4(m.emission[0], m.emission[1], m.emission[2], 0.f);
  }
  for (size_t i = 0; i < n_lights; ++i) {
    const rt_point_light& l = lights[i];
    lts[2 * i + 0] = make_float4(l.position[0], l.position[1], l.position[2], 0.f);
    lts[2 * i + 1] = make_float4(l.intensity[0], l.intensity[1], l.intensity[2], 0.f);
  }
  // primitives whose material emits (Eq. 7's L_e), sampled as lights, in id order
  std::vector<int> emit;
  auto emits = [&](uint32_t m) {
    const float* e = materials[m].emission;
    return std::max(e[0], std::max(e[1], e[2])) > 0.f;
  };
  for (size_t i = 0; i < n_spheres; ++i)
    if (emits(spheres[i].material)) emit.push_back((int)i);
  for (size_t i = 0; i < n_triangles; ++i)
    if (emits(triangles[i].material)) emit.push_back((int)(n_spheres + i));
  s->n_emitters = (int64_t)emit.size();
  size_t np = (size_t)s->n_prims;
  if ((st = ensure(s->raw_sph, n_spheres * sizeof(rt_sphere))) ||
      (st = ensure(s->emitters, std::max<size_t>(emit.size(), 1) * sizeof(int))) ||
      (st = ensure(s->raw_tri, n_triangles * sizeof(rt_triangle))) ||
      (st = ensure(s->prims_id, np * 48)) || (st = ensure(s->prims_leaf, np * 48)) ||
      (st = ensure(s->mats, mats.size() * 16)) || (st = ensure(s->lights, lts.size() * 16))) {
    rt_scene_destroy(s);
    return st;
  }
  cudaError_t e = cudaMalloc(&s->status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(s->status, 0, sizeof(unsigned));
  if (e == cudaSuccess && n_spheres)
    e = cudaMemcpy(s->raw_sph.p, spheres, n_spheres * sizeof(rt_sphere), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_triangles)
    e = cudaMemcpy(s->raw_tri.p, triangles, n_triangles * sizeof(rt_triangle), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->mats.p, mats.data(), mats.size() * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->lights.p, lts.data(), lts.size() * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !emit.empty())
    e = cudaMemcpy(s->emitters.p, emit.data(), emit.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    rt_scene_destroy(s);
    return cuda_error(e, "rt_scene_create upload");
  }
  if ((st = pack(s, 0)) != RT_OK) {
    rt_scene_destroy(s);
    return st;
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    rt_scene_destroy(s);
    return cuda_error(e, "rt_scene_create");
  }
  *out = s;
  return RT_OK;
}

rt_status rt_scene_set_area_lights(rt_scene* s, const rt_area_light* lights, size_t n) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_scene_set_area_lights: scene is NULL");
  if (n && !lights) return set_error(RT_ERR_INVALID_ARG, "rt_scene_set_area_lights: NULL array with n > 0");
  if (n > (1u << 20)) return set_error(RT_ERR_UNSUPPORTED, "rt_scene_set_area_lights: more than 2^20 lights");
  std::vector<float4> rec(4 * (n ? n : 1));
  for (size_t i = 0; i < n; ++i) {
    const rt_area_light& a = lights[i];
    if (!finite3(a.corner) || !finite3(a.edge_u) || !finite3(a.edge_v) || !finite3(a.radiance) ||
        a.radiance[0] < 0.f || a.radiance[1] < 0.f || a.radiance[2] < 0.f)
      return set_error(RT_ERR_INVALID_ARG, "rt_scene_set_area_lights: non-finite value or negative radiance");
    // normal and area from edge_u x edge_v (host FP64, stored in FP32)
    double cx = (double)a.edge_u[1] * a.edge_v[2] - (double)a.edge_u[2] * a.edge_v[1];
    double cy = (double)a.edge_u[2] * a.edge_v[0] - (double)a.edge_u[0] * a.edge_v[2];
    double cz = (double)a.edge_u[0] * a.edge_v[1] - (double)a.edge_u[1] * a.edge_v[0];
    double area = std::sqrt(cx * cx + cy * cy + cz * cz);
    if (!(area > 0.0) || !std::isfinite(area))
      return set_error(RT_ERR_INVALID_ARG, "rt_scene_set_area_lights: degenerate parallelogram");
    rec[4 * i + 0] = make_float4(a.corner[0], a.corner[1], a.corner[2], (float)area);
    rec[4 * i + 1] = make_float4(a.edge_u[0], a.edge_u[1], a.edge_u[2], (float)(cx / area));
    rec[4 * i + 2] = make_float4(a.edge_v[0], a.edge_v[1], a.edge_v[2], (float)(cy / area));
    rec[4 * i + 3] = make_float4(a.radiance[0], a.radiance[1], a.radiance[2], (float)(cz / area));
  }
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return cuda_error(e, "rt_scene_set_area_lights");
  rt_status st = ensure(s->alights, rec.size() * 16);
  if (st) return st;
  // the frames already queued on any stream may still read the old lights
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(s->alights.p, rec.data(), rec.size() * 16, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "rt_scene_set_area_lights");
  s->n_alights = (int64_t)n;
  return RT_OK;
}

rt_status rt_scene_update(rt_scene* s, const rt_sphere* spheres, const rt_triangle* triangles, void* stream) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_scene_update: scene is NULL");
  if ((s->n_spheres && !spheres) || (s->n_tris && !triangles))
    return set_error(RT_ERR_INVALID_ARG, "rt_scene_update: NULL array with a non-zero count");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  // host or device source: the copy direction follows from the pointers
  if (s->n_spheres)
    e = cudaMemcpyAsync(s->raw_sph.p, spheres, s->n_spheres * sizeof(rt_sphere), cudaMemcpyDefault, st);
  if (e == cudaSuccess && s->n_tris)
    e = cudaMemcpyAsync(s->raw_tri.p, triangles, s->n_tris * sizeof(rt_triangle), cudaMemcpyDefault, st);
  if (e != cudaSuccess) return cuda_error(e, "rt_scene_update");
  s->built = false;
  return pack(s, st);
}

rt_status rt_scene_sync(rt_scene* s, void* stream) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_scene_sync: scene is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  rt_status rs = issue_pending_copy(s);   // the last rt_render_host_async frame's image
  if (rs) return rs;
  cudaError_t e = cudaStreamSynchronize(st);
  // and the host copies of rt_render_host_async, which follow the stream's frames
  if (e == cudaSuccess && s->copy_stream) e = cudaStreamSynchronize(s->copy_stream);
  if (e != cudaSuccess) return cuda_error(e, "rt_scene_sync");
  unsigned flags = 0;
  e = cudaMemcpy(&flags, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "rt_scene_sync status");
  if (flags) {
    cudaMemset(s->status, 0, sizeof(unsigned));
    if (flags & kErrQueueOverflow)
      return set_error(RT_ERR_QUEUE_OVERFLOW, "a ray queue overflowed; rays were dropped (raise queue_capacity)");
    if (flags & kErrBadTree) return set_error(RT_ERR_CUDA, "traversal met a link outside the BVH arrays");
    if (flags & kErrBadMaterial)
      return set_error(RT_ERR_INVALID_ARG, "rt_scene_update: a material index out of range (material 0 used)");
    if (flags & kErrNrcTimeout) return set_error(RT_ERR_CUDA, "a radiance-cache tensor-core wait timed out");
    if (flags & kErrTraversalLimit)
      return set_error(RT_ERR_TRAVERSAL_LIMIT, "a ray reached the traversal step cap or the stack depth");
  }
  return RT_OK;
}

}  // extern "C"
