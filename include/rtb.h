/*
 * rtb.h - C ABI of the B300 (sm_103a) Whitted ray tracer, librtb.so.
 *
 * The method is that of "Massively Parallel Ray Tracing Algorithm Using GPU"
 * (Qin, Lin, Huang): one thread per ray, the recursion over reflection /
 * refraction turned into an iteration whose trip count is the recursion
 * depth (Sec. IV.A), one shadow ray per light at every hit (Alg. 1), the
 * ray-sphere quadratic of Eq. 9-12 and shading from Eq. 6-8.  Triangles, the
 * BVH and the wavefront queues extend it.
 *
 * Conventions shared by every call:
 *   - Primitive ids: sphere i -> i, triangle j -> n_spheres + j; -1 = miss.
 *   - Images are H x W x 3 float32, row-major, row 0 at the top.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Calls are stream-ordered.  Argument errors are returned at once.
 *     Errors raised inside kernels (queue overflow, traversal limit) are
 *     latched in the scene and returned by the next rt_scene_sync (or by
 *     rt_render_ex when it is given a stats pointer, which syncs).
 *   - rt_last_error() gives a message for the last non-OK status of the
 *     calling thread.
 *   - Host arrays passed in are copied; the caller keeps ownership.  Device
 *     buffers passed in (out_rgb, AOVs, ray arrays) are owned by the caller
 *     and must stay alive until the stream reaches the call.
 */
#ifndef RTB_H
#define RTB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTB_ABI_VERSION 1
#define RT_MAX_DEPTH 16

typedef enum rt_status {
  RT_OK = 0,
  RT_ERR_INVALID_ARG = 1,     /* bad pointer, size, NaN/Inf, radius <= 0, bad material index ... */
  RT_ERR_OOM = 2,             /* a device or pinned allocation failed */
  RT_ERR_CUDA = 3,            /* any other CUDA runtime error */
  RT_ERR_NOT_BUILT = 4,       /* BVH traversal requested before rt_bvh_build */
  RT_ERR_QUEUE_OVERFLOW = 5,  /* a ray queue was full: rays were dropped */
  RT_ERR_TRAVERSAL_LIMIT = 6, /* a ray hit the traversal step cap or the stack depth */
  RT_ERR_UNSUPPORTED = 7      /* a valid request this build does not handle */
} rt_status;

/* Sphere of Eq. 9: |p - center|^2 = radius^2.  radius > 0. */
typedef struct rt_sphere {
  float center[3];
  float radius;
  uint32_t material;          /* index into the material array */
} rt_sphere;

/* Triangle (v0, v1, v2); two-sided; its geometric normal is
 * normalize((v1-v0) x (v2-v0)).  Degenerate triangles are never hit. */
typedef struct rt_triangle {
  float v0[3], v1[3], v2[3];
  uint32_t material;
} rt_triangle;

enum { RT_MAT_DIFFUSE = 0, RT_MAT_MIRROR = 1, RT_MAT_DIELECTRIC = 2 };

/* Surface model (the f_r and L_e of Eq. 7-8):
 *   DIFFUSE    : Lambert (albedo) + Phong (ks, shininess); reflectivity ignored.
 *   MIRROR     : (1 - reflectivity) x the DIFFUSE local term, plus a
 *                reflection ray of weight reflectivity.
 *   DIELECTRIC : no local term; Fresnel-Schlick reflection ray (weight R)
 *                and Snell refraction ray (weight 1 - R; none on total
 *                internal reflection); index of refraction `ior`.
 *   emission   : L_e, added at every hit.  A primitive whose material
 *                emits (some channel > 0) is also a light: each pass
 *                samples one point of it per shaded vertex, like an area
 *                light (triangles emit on both faces). */
typedef struct rt_material {
  uint32_t kind;
  float albedo[3];
  float ks;
  float shininess;
  float reflectivity;
  float ior;
  float emission[3];
} rt_material;

/* Point light: no distance fall-off; intensity per channel. */
typedef struct rt_point_light {
  float position[3];
  float intensity[3];
} rt_point_light;

/* Pinhole camera, vertical field of view in degrees, aspect W/H,
 * pixel centres at +0.5. */
typedef struct rt_camera {
  float eye[3], look_at[3], up[3];
  float vfov_deg;
} rt_camera;

enum {
  RT_FLAG_STAGE_TIMING = 1,   /* record per-stage CUDA events (stats.ms_*) */
  RT_FLAG_COUNT_WORK = 2,     /* count node visits / primitive tests (slower kernels) */
  RT_FLAG_NO_GRAPH = 4,       /* launch the kernels directly, no CUDA graph */
  RT_FLAG_PER_DEPTH_WAVEFRONT = 8, /* queue every depth (default: depths 0 and 1 as wavefronts,
                                      deeper rays depth first, one lane per path segment) */
  RT_FLAG_DIFFUSE_BOUNCE = 16,     /* Monte-Carlo GI (Eq. 8's hemisphere integral): below the
                                      last depth, every non-dielectric hit with reflectivity < 1
                                      and some albedo > 0 also sends one cosine-weighted ray of
                                      weight pi (1 - reflectivity) albedo (f_r = albedo, as in the
                                      light terms), drawn from the pass (rt_pass).  That ray adds
                                      no emission where it hits: emitters are sampled as lights.
                                      Only the Lambert lobe is integrated.  Such a frame runs
                                      every depth as a wavefront (as RT_FLAG_PER_DEPTH_WAVEFRONT).
                                      With the radiance cache: frames and passes take it (the
                                      cache then learns from GI paths); a batch does not
                                      (RT_ERR_UNSUPPORTED). */
  RT_FLAG_SERIAL_STAGES = 64,      /* run each depth's shadow kernel on the caller's stream after
                                      that depth's closest-hit kernel, not beside the next depth on
                                      a side stream: with RT_FLAG_STAGE_TIMING every kernel is then
                                      timed alone (a measurement mode; frames take longer) */
  RT_FLAG_DETERMINISTIC = 32       /* accumulate every pixel in 64-bit fixed point (units of
                                      2^-32, contributions clamped to +-2^30) with integer
                                      atomics, whose sum does not depend on the order the rays
                                      finish in, and convert to float32 at the end of the frame:
                                      the image is bit-identical from run to run.  Costs a
                                      scene-owned buffer of 24 bytes a pixel and one conversion
                                      pass.  Not with the radiance cache or a batch
                                      (RT_ERR_UNSUPPORTED). */
};

typedef struct rt_render_options {
  int32_t use_bvh;            /* 1: BVH traversal; 0: test every primitive (Alg. 1's loop) */
  int32_t flags;              /* RT_FLAG_* */
  float background[3];        /* radiance of a miss */
  float eps_scale;            /* origin offset eps = eps_scale * max(1, |p|_inf) */
  int64_t queue_capacity;     /* rays per secondary / shadow queue; 0 = default */
  int64_t traversal_cap;      /* loop steps per ray before RT_ERR_TRAVERSAL_LIMIT; 0 = default */
  uint32_t* ray_counts;       /* NULL, or a device buffer of H*W*2*(max_depth+1) uint32 that a frame
                                 rendered with RT_FLAG_COUNT_WORK clears and fills: for pixel p and
                                 depth d, [p][d][0] = closest-hit rays traced at depth d and
                                 [p][d][1] = shadow rays cast from its depth-d hits (the per-pixel
                                 split of rt_render_stats' rays_per_depth and shadow_per_depth).
                                 The radiance cache's training rays are not counted.  Frames only
                                 (rt_render_ex, rt_render_pass, rt_render_nrc); a batch ignores it. */
} rt_render_options;

/* Defaults: use_bvh 1, flags 0, background 0.1, eps_scale 1e-4,
 * queue_capacity max(2*W*H, 65536) closest-hit rays (shadow queue:
 * n_lights x that), traversal_cap 4 * nodes + 64, ray_counts NULL. */
void rt_render_options_default(rt_render_options* opt);

typedef struct rt_render_stats {
  uint64_t primary, shadow, secondary;           /* rays traced per class */
  uint64_t rays_per_depth[RT_MAX_DEPTH + 1];     /* closest-hit rays at depth d */
  uint64_t shadow_per_depth[RT_MAX_DEPTH + 1];   /* shadow rays cast from depth-d hits */
  uint64_t hits_per_depth[RT_MAX_DEPTH + 1];
  uint64_t node_visits[2], prim_tests[2];        /* [closest, any]; RT_FLAG_COUNT_WORK only */
  uint64_t node_visits_per_depth[2][RT_MAX_DEPTH + 1];  /* same, per depth */
  uint32_t max_visits_per_depth[2][RT_MAX_DEPTH + 1];   /* most node visits of one ray */
  float ms_total;                                /* RT_FLAG_STAGE_TIMING only */
  float ms_trace;                                /* closest-hit + shade kernels (sum of their times) */
  float ms_shadow;                               /* any-hit kernels; they overlap the next depth's trace */
  int32_t launches;                              /* kernels this render launched */
  uint64_t box_tests[2];                         /* child boxes tested ([closest, any]; RT_FLAG_COUNT_WORK only);
                                                    node_visits counts 4-wide nodes, each testing 2 to 4 boxes */
} rt_render_stats;

typedef struct rt_bvh_info {
  int64_t n_prims;
  int64_t n_nodes;            /* internal nodes reachable from the root */
  int64_t root;               /* index of the root node in the exported layout */
  int32_t max_depth;          /* deepest leaf (root = 0) */
  int32_t max_leaf_size;
  double sah_cost;            /* SAH cost (C_trav = C_isect = 1) of the tree */
  double sah_cost_lbvh;       /* same, of the plain LBVH before refinement */
  float build_ms;             /* last build, when timed */
  int32_t build_launches;     /* kernels (and memsets) the last build issued */
} rt_bvh_info;

typedef struct rt_scene rt_scene;

int rt_abi_version(void);
const char* rt_last_error(void);

/* A parallelogram light: the points corner + a edge_u + b edge_v, a and b
 * in [0, 1].  It emits `radiance` (per channel, >= 0) on the side of
 * edge_u x edge_v only, and is not geometry: rays do not hit it.  Each
 * pass samples one point of it per shaded vertex (see rt_render_pass). */
typedef struct rt_area_light {
  float corner[3], edge_u[3], edge_v[3];
  float radiance[3];
} rt_area_light;

/* One pass of a progressive render (Sec. IV.A: the paper samples each light
 * once per pass and lets the image converge over passes).  The random
 * numbers of pass `index` come from Philox4x32-10 keyed by `seed` and
 * counted by (pixel, index, path vertex, slot); a sample is stratified over
 * strata x strata consecutive passes.  jitter != 0 moves each camera ray to
 * a sampled point inside its pixel (anti-aliasing); otherwise it goes
 * through the pixel centre.  rt_render and rt_render_ex render pass
 * {seed 0, index 0, strata 1, no jitter}. */
typedef struct rt_pass {
  uint64_t seed;
  int32_t index;    /* >= 0 */
  int32_t strata;   /* >= 1 */
  int32_t jitter;
  int32_t reserved; /* 0 */
} rt_pass;

/* The scene of the paper's problem statement (Sec. II; Sec. IV.B): the
 * objects - spheres of Eq. 9, plus triangles - with their materials (the
 * f_r and L_e of Eq. 6-8) and the point lights that Alg. 1 casts shadow
 * rays to.
 * Copies the host arrays to the device and packs them into the device
 * layout.  Spheres and triangles may be empty (not both NULL with n > 0).
 * Validates every value: RT_ERR_INVALID_ARG on NaN/Inf, radius <= 0 or a
 * material index >= n_materials.  Synchronous. */
rt_status rt_scene_create(const rt_sphere* spheres, size_t n_spheres, const rt_triangle* triangles,
                          size_t n_triangles, const rt_material* materials, size_t n_materials,
                          const rt_point_light* lights, size_t n_lights, rt_scene** out);

/* Replaces the scene's area lights (n may be 0).  RT_ERR_INVALID_ARG on a
 * non-finite value, a negative radiance or a degenerate parallelogram.
 * Synchronous: waits for the device. */
rt_status rt_scene_set_area_lights(rt_scene* s, const rt_area_light* lights, size_t n);

/* Replaces the geometry with new arrays of the same counts (a moving
 * scene).  The arrays may live in host memory (pinned memory makes the
 * copy asynchronous) or in device memory; the copy and the on-device
 * repacking run on `stream`.  The BVH must be rebuilt afterwards.
 * Values are not validated (use rt_scene_create for checked input),
 * except material indices: one out of range is replaced by material 0 and
 * reported by the next rt_scene_sync (RT_ERR_INVALID_ARG).  The emissive
 * primitives sampled as lights are those that rt_scene_create found: an
 * update that changes a primitive's material changes its shading only. */
rt_status rt_scene_update(rt_scene* s, const rt_sphere* spheres, const rt_triangle* triangles,
                          void* stream);

/* The acceleration structure, which the paper names only among the
 * speed-ups of Sec. II (its Alg. 1 tests every object, which use_bvh = 0
 * keeps); the result is the same nearest hit.
 * Builds the BVH on the device: 30-bit Morton codes, radix sort (by the
 * codes' top 24 bits for at most 2^17 primitives, else all 30), LBVH
 * hierarchy, bottom-up boxes, binned-SAH rebuild of the top levels and
 * SAH leaf collapsing.  Stream-ordered; rebuild allowed at any time. */
rt_status rt_bvh_build(rt_scene* s, void* stream);

/* Fills *info (syncs the stream). */
rt_status rt_bvh_get_info(rt_scene* s, rt_bvh_info* info, void* stream);

/* Copies the binary BVH to host buffers (syncs), for inspection.
 * nodes: n_nodes x 16 floats per node: child 0's lo.x, hi.x, lo.y, hi.y;
 * child 1's lo.x, hi.x, lo.y, hi.y; lo.z, hi.z of child 0 then of child 1;
 * two int32 child links (>= 0: node index; < 0: leaf ~(start << 3 |
 * count - 1) over prim_order positions); two unused words.  prim_order:
 * n_prims int32 (leaf order -> primitive id); morton: n_prims uint32
 * sorted codes, in leaf order, with the bits below the sort key cleared (the
 * low 6 bits for at most 2^17 primitives, none above).  Any pointer may be
 * NULL. */
rt_status rt_bvh_export(rt_scene* s, float* nodes, int64_t nodes_capacity, int32_t* prim_order,
                        uint32_t* morton, void* stream);

/* Copies the 4-wide tree that the traversal kernels walk to a host buffer
 * (syncs), for inspection.  Node i is 32 floats: lo.x[4], hi.x[4], lo.y[4],
 * hi.y[4], lo.z[4], hi.z[4], then four int32 child links (>= 0: node
 * index; < 0 and not INT32_MIN: leaf ~(start << 3 | count - 1) over
 * prim_order positions; INT32_MIN: unused slot, box lo = +inf, hi = -inf),
 * then the number of used slots and three unused words.  There is one
 * node per binary node slot, at the binary node's index; the root is the
 * root that rt_bvh_get_info reports, and nodes that cannot be reached from
 * it hold data that is never read.  Writes min(capacity, slots) nodes;
 * *n_nodes (if not NULL) receives the number of slots.  The 4-wide nodes
 * are a device layout of this library: the paper's tree is binary
 * (rt_bvh_export). */
rt_status rt_bvh_export_wide(rt_scene* s, float* nodes, int64_t nodes_capacity, int64_t* n_nodes, void* stream);

/* One pass of a progressive render: renders pass `pass->index` (with the
 * options and limits of rt_render_ex) and folds it into accum_rgb_device
 * (H*W*3 float32), the running mean of passes 0..index: pass 0 overwrites
 * it, pass k adds (image - accum) / (k + 1).  Passes of one image must run
 * in order on one stream.  stats (nullable) receives the pass's ray counts
 * as rt_render_ex's do (syncs the stream). */
rt_status rt_render_pass(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth,
                         const rt_pass* pass, float* accum_rgb_device, const rt_render_options* options,
                         rt_render_stats* stats, void* stream);

/* One frame of the paper's method (Sec. IV.A; Alg. 1; Eq. 6-12): a camera
 * ray per pixel, its closest hit (spheres by Eq. 9-12, triangles by
 * Moller-Trumbore), local shading by Eq. 6-8 with one shadow ray per point
 * light (Alg. 1), the reflection / refraction recursion (Fig. 3) turned into
 * an iteration over depths 0..max_depth (Sec. IV.A), and every
 * contribution added onto its pixel (Sec. IV.A).
 * Renders into out_rgb_device (H*W*3 float32, overwritten; caller-owned).
 * RT_ERR_INVALID_ARG on a NULL scene or image, an invalid camera, a size
 * < 1 or max_depth outside [0, RT_MAX_DEPTH]; RT_ERR_NOT_BUILT before
 * rt_bvh_build; kernel errors are latched (rt_scene_sync). */
rt_status rt_render(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth,
                    float* out_rgb_device, void* stream);

/* rt_render (the frame of Sec. IV.A, Alg. 1, Eq. 6-12) with options
 * (NULL = defaults; use_bvh = 0 is Alg. 1's loop over every object),
 * optional primary-ray AOVs (device, H*W: hit primitive id / hit distance,
 * inf on a miss) and optional stats (host; filled after a stream sync, which
 * also returns the latched kernel errors).
 *
 * CUDA graphs: once a scene has been built and rendered at a given size,
 * depth and options, rt_scene_update from device arrays, rt_bvh_build and
 * rt_render / rt_render_ex without stats allocate nothing and never wait
 * for the host, so a frame's calls can be captured into a CUDA graph
 * (stream capture on `stream`) and replayed.  A replay repeats the captured
 * camera and sizes, and reads the geometry arrays anew. */
rt_status rt_render_ex(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth,
                       float* out_rgb_device, const rt_render_options* opt, int32_t* aov_prim,
                       float* aov_t, rt_render_stats* stats, void* stream);

/* Stage times (ms) of the last frame rendered with RT_FLAG_STAGE_TIMING,
 * from CUDA events recorded on its stream: the whole frame, the
 * closest-hit + shade kernels and the shadow kernels.  Waits for that
 * frame's last event only. */
rt_status rt_render_stage_times(rt_scene* s, float* ms_total, float* ms_trace, float* ms_shadow);

/* rt_render into a HOST buffer: renders into scene-owned device memory,
 * copies back on `stream` and waits for it. */
rt_status rt_render_host(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth,
                         float* out_rgb_host, const rt_render_options* opt, void* stream);

/* rt_render_host for a stream of frames: returns once the frame is queued.
 * The frame renders on `stream` into one of two scene-owned device images
 * (alternating from call to call; a frame waits for the copy that last used
 * its image) and is copied to out_host (H*W*3 float32; pinned memory for an
 * asynchronous copy) on a copy stream of the scene.  The copy is queued by
 * the next call, after the work already queued on its stream (the next
 * frame's update and build), so that it runs beside the next frame's
 * render; or by rt_scene_sync.  out_host is complete, and may be reused,
 * once rt_scene_sync(s, stream) has returned, which also waits for the copy
 * stream.  Errors as rt_render_ex. */
rt_status rt_render_host_async(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth,
                               float* out_host, const rt_render_options* options, void* stream);

/* The primary rays rt_render traces (device arrays, H*W*3 float each,
 * pixel-major): the same device function generates them. */
rt_status rt_camera_rays(const rt_camera* cam, int width, int height, float* o_device,
                         float* d_device, void* stream);

/* The closest-hit query of the frame (Eq. 9-12 for spheres, Alg. 1's
 * nearest object) on caller rays.
 * Closest hit for n rays (device arrays n*3 float), t in (tmin, inf):
 * prim id (or -1) and t (inf on a miss).  use_bvh as in the options. */
rt_status rt_trace_closest(rt_scene* s, const float* o_device, const float* d_device, int64_t n,
                           float tmin, int use_bvh, int32_t* prim_device, float* t_device,
                           void* stream);

/* Alg. 1's shadow test on caller rays: any hit with t in (tmin, tmax[i])
 * for n rays: occluded[i] = 0/1. */
rt_status rt_trace_any(rt_scene* s, const float* o_device, const float* d_device,
                       const float* tmax_device, int64_t n, float tmin, int use_bvh,
                       uint8_t* occluded_device, void* stream);

/* Limits of rt_render_noalloc's fixed scratch array. */
#define RT_NOALLOC_MAX_PIXELS 16384
#define RT_NOALLOC_MAX_LIGHTS 4

/* rt_render without any device allocation, for callers that may not call
 * cudaMalloc while they render (a host application or plug-in framework
 * that owns the GPU memory budget and forbids allocation after start-up,
 * or code confined to a pre-reserved pool).  The paper has no counterpart:
 * this is a deployment variant of rt_render.
 *   - Same frame as rt_render with default options (BVH traversal,
 *     background 0.1, eps_scale 1e-4); the scene must be built.
 *   - Ray queues and counters live in one file-scope device array of
 *     about 9.4 MB (counters + 2 x 2*RT_NOALLOC_MAX_PIXELS ray records +
 *     2*RT_NOALLOC_MAX_PIXELS*RT_NOALLOC_MAX_LIGHTS shadow records, 48 B
 *     each) that every GPU loading the library holds until the process
 *     exits.  width*height > RT_NOALLOC_MAX_PIXELS or more than
 *     RT_NOALLOC_MAX_LIGHTS lights (point lights, area lights and
 *     emissive primitives together) -> RT_ERR_UNSUPPORTED with a message.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first
 *     call before any stream capture.
 *   - All calls share the one array (the counters are cleared at the start
 *     of each call): calls whose work overlaps on the GPU - on different
 *     streams, or from different threads - race and corrupt each other.
 *     Serialise them on one stream.
 *   - Queue overflow (many dielectric bounces) is latched like rt_render's
 *     and returned by rt_scene_sync. */
rt_status rt_render_noalloc(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth,
                            float* out_rgb_device, void* stream);

/* ---- neural radiance cache (no counterpart in the paper) -------------
 * A small MLP that stands in for the rest of a path after a fixed bounce:
 * 81 features (normalised hit position, normal, view direction and sin/cos
 * of 2^k pi x for k = 0..11) -> 64 -> 64 -> 64 -> 64 -> 3, ReLU hidden
 * layers, exp output; BF16 weights and activations with FP32 accumulation
 * on the tensor cores; trained online with Adam (FP32 master weights) on
 * the relative-L2 loss mean((y - t)^2 / (y^2 + 0.01)) against the radiance
 * the tracer computes for a seeded subset of the cached hits. */
typedef struct rt_nrc rt_nrc;

typedef struct rt_nrc_config {
  int32_t train_batch;        /* training samples per frame (default 65536) */
  int32_t terminate_depth;    /* depth whose hits read the cache (default 2) */
  float lr, beta1, beta2, eps;/* Adam (1e-2, 0.9, 0.99, 1e-8) */
  uint64_t seed;              /* weight initialisation and sample selection */
} rt_nrc_config;

#define RT_NRC_PARAMS 18883   /* W0[64][96] W1..W3[64][64] W4[3][64], b0..b3[64], b4[3] (FP32) */

void rt_nrc_config_default(rt_nrc_config* cfg);
/* He-uniform initial weights (seeded), zero biases; the encoding normalises
 * positions by the scene's bounding box. */
rt_status rt_nrc_create(rt_scene* s, const rt_nrc_config* cfg, rt_nrc** out);
rt_status rt_nrc_destroy(rt_nrc* nrc);
/* FP32 master parameters, RT_NRC_PARAMS floats (layout above); set also
 * resets the Adam moments and step. */
rt_status rt_nrc_get_params(rt_nrc* nrc, float* host_params, void* stream);
rt_status rt_nrc_set_params(rt_nrc* nrc, const float* host_params, void* stream);
/* Writes the cache to a file: its configuration, FP32 parameters, Adam
 * moments and step (little-endian, behind a magic tag and a format
 * version).  Syncs the stream.  RT_ERR_INVALID_ARG when the file cannot
 * be written. */
rt_status rt_nrc_save(rt_nrc* nrc, const char* path, void* stream);
/* Restores a cache written by rt_nrc_save into nrc: parameters, Adam
 * moments, step and configuration (the encoding box stays that of nrc's
 * scene).  Syncs the stream.  RT_ERR_INVALID_ARG on a missing or truncated
 * file, another format, or an invalid configuration or non-finite value;
 * nrc is then unchanged. */
rt_status rt_nrc_load(rt_nrc* nrc, const char* path, void* stream);
/* Gradient of the last training step (RT_NRC_PARAMS floats) and its loss. */
rt_status rt_nrc_get_grads(rt_nrc* nrc, float* host_grads, float* host_loss, void* stream);
/* exp(MLP(encode(p, n, v))) for n hits given as n x 9 device floats (p, n, v);
 * out: n x 3 device floats. */
rt_status rt_nrc_infer(rt_nrc* nrc, rt_scene* s, const float* pnv_device, int64_t n, float* out_device,
                       void* stream);
/* One training step (gradient + Adam) on n samples: pnv n x 9, target n x 3. */
rt_status rt_nrc_train_step(rt_nrc* nrc, rt_scene* s, const float* pnv_device, const float* target_device,
                            int64_t n, void* stream);
/* A frame whose hits at cfg.terminate_depth take the radiance they reflect
 * from the cache (no shadow or secondary rays there; the hit's own emission
 * L_e is added as at any hit, unless a diffuse bounce reached it); when
 * `train` is set, a seeded subset of those hits (about train_batch) is also
 * traced to max_depth with unit weight, the results become training targets
 * and one Adam step runs after the frame.  Options (NULL = defaults) and stats as in rt_render_ex
 * (rays actually traced). */
rt_status rt_render_nrc(rt_scene* s, rt_nrc* nrc, const rt_camera* cam, int width, int height, int max_depth,
                        float* out_rgb_device, int train, const rt_render_options* opt, rt_render_stats* stats,
                        void* stream);

/* rt_render_pass with the radiance cache: pass `pass->index` (its light
 * samples, jitter and, with RT_FLAG_DIFFUSE_BOUNCE, its bounce directions)
 * rendered as rt_render_nrc renders a frame - hits at the cache's depth take
 * the radiance they reflect from the cache, a seeded subset is traced on
 * into training targets when `train` is set, then one training step - and
 * folded into accum_rgb_device as rt_render_pass does.  With the diffuse
 * bounce the training targets are Monte-Carlo GI paths (Eq. 8's hemisphere
 * integral), and the frame runs every depth as a wavefront.  The cache has
 * no counterpart in the paper; the passes are those of Sec. IV.A. */
rt_status rt_render_nrc_pass(rt_scene* s, rt_nrc* nrc, const rt_camera* cam, int width, int height, int max_depth,
                             const rt_pass* pass, float* accum_rgb_device, int train,
                             const rt_render_options* options, rt_render_stats* stats, void* stream);

/* ---------------------------------------------------------------------------
 * Batched rendering.  The paper renders one scene at a time; this renders
 * many scenes of uneven size and resolution in one persistent launch
 * (replayed from a CUDA graph), each with its own BVH, camera and image.
 * A warp takes a tile of 32 pixels of one scene and carries every ray it
 * spawns (shadow rays, reflections, refractions; Sec. IV.A, Alg. 1) to
 * max_depth depth first, sharing pending rays among its lanes; then it
 * takes the next tile of any scene.  The image is the one rt_render makes.
 * ------------------------------------------------------------------------- */
typedef struct rt_tune {
  int32_t tile_w, tile_h;   /* pixels of a warp's tile; tile_w * tile_h == 32 */
  int32_t block_threads;    /* threads a block: 64, 128 or 256 */
  int32_t blocks_per_sm;    /* persistent grid, blocks per SM; 0 = as many as fit */
} rt_tune;

typedef struct rt_batch rt_batch;

/* A batch of n >= 1 frames: frame i renders scenes[i] (the same scene may
 * appear more than once, e.g. several views) seen by cameras[i] at
 * widths[i] x heights[i] into out_rgb[i] (caller-owned device buffers,
 * H*W*3 float32, overwritten).  Copies the arrays (host); the scenes must
 * outlive the batch and have a BVH when it renders.  options: NULL =
 * defaults; use_bvh must be set.  RT_ERR_INVALID_ARG on a NULL argument,
 * n < 1, a size < 1, an invalid camera or max_depth outside
 * [0, RT_MAX_DEPTH]. */
rt_status rt_batch_create(rt_scene* const* scenes, int32_t n, const rt_camera* cameras, const int32_t* widths,
                          const int32_t* heights, int32_t max_depth, float* const* out_rgb,
                          const rt_render_options* options, rt_batch** out);
/* n cameras (host array), used from the next rt_batch_render on. */
rt_status rt_batch_set_cameras(rt_batch* b, const rt_camera* cameras);
/* Renders every frame of the batch on `stream` (one kernel, from a CUDA
 * graph that is captured once per tune).  tune: NULL = the last autotuned
 * choice, else a default.  stats (nullable): summed over the frames; asking
 * for them syncs the stream and returns the scenes' latched errors. */
rt_status rt_batch_render(rt_batch* b, const rt_tune* tune, rt_render_stats* stats, void* stream);
/* Times candidate tunes on this batch (each rendered 3 times, CUDA events
 * on `stream`) and keeps the fastest for rt_batch_render(b, NULL, ...).
 * best and best_ms are nullable.  Renders the batch (the images are left
 * valid). */
rt_status rt_batch_autotune(rt_batch* b, rt_tune* best, float* best_ms, void* stream);
rt_status rt_batch_destroy(rt_batch* b);

/* The radiance cache (rt_nrc) inside the batch's persistent launch: every
 * frame's hits at the cache's terminate_depth end their path in the cache
 * (one inference record each, the network's answer added after the launch);
 * with train set, a seeded subset of them (about train_batch over the whole
 * batch) is traced on to max_depth with unit weight into training targets,
 * and one training step runs after the launch.  Every frame must show the
 * scene the cache was created for (RT_ERR_INVALID_ARG otherwise); not with
 * RT_FLAG_DIFFUSE_BOUNCE (RT_ERR_UNSUPPORTED).  Launched directly (no
 * graph): the batch kernel, the inference kernel, and with train the
 * training, Adam and repack kernels.  tune: NULL = the batch's autotuned
 * choice.  stats as rt_batch_render.  The paper has no counterpart: it
 * neither batches nor caches (Sec. IV.A per frame). */
rt_status rt_batch_render_nrc(rt_batch* b, rt_nrc* nrc, int train, const rt_tune* tune, rt_render_stats* stats,
                              void* stream);

/* The one-call form of a batch: renders frame i = (scenes[i], cameras[i],
 * widths[i] x heights[i]) into out_rgb[i] for i < n, to max_depth, in one
 * persistent launch, with `tune` (NULL = a default tile and block shape)
 * and default options.  It creates a batch, renders it, waits for `stream`
 * and destroys the batch, so it pays the graph capture every call; a
 * caller that renders the same frames again keeps an rt_batch instead.
 * Errors as rt_batch_create and rt_batch_render, and the scenes' latched
 * kernel errors.  Batching has no counterpart in the paper. */
rt_status rt_render_batch(rt_scene* const* scenes, const rt_camera* cameras, const int32_t* widths,
                          const int32_t* heights, int32_t n, int32_t max_depth, float* const* out_rgb,
                          const rt_tune* tune, void* stream);

/* A measurement helper with no counterpart in the paper: the L2 read
 * bandwidth of the current device in GB/s, the roofline of traversal
 * kernels whose nodes and primitives fit in L2.  Allocates a device buffer
 * of `bytes` (64 KB .. 2 GB; below the L2's size to measure L2), reads it
 * once to bring it into L2, then times `reps` more streaming reads that
 * bypass L1 (CUDA events on `stream`), frees it and returns the bytes read
 * per second.  Synchronous. */
rt_status rt_probe_l2_read(size_t bytes, int reps, float* gbs, void* stream);

/* Waits for `stream` (and for the host copies of rt_render_host_async)
 * and returns (and clears) the latched kernel error.  Host-side plumbing:
 * no counterpart in the paper. */
rt_status rt_scene_sync(rt_scene* s, void* stream);

/* Waits for the device and frees everything the scene owns (NULL is a
 * no-op).  Host-side plumbing: no counterpart in the paper. */
rt_status rt_scene_destroy(rt_scene* s);

#ifdef __cplusplus
}
#endif
#endif /* RTB_H */
